// The real sine transform variant of the analysis (Sec. 4: the real sine FFT leaves the boundary
// unchanged).  The orthonormal type-I sine transform of the interior of a grid of ny x nx nodes is,
// exactly, the unitary DFT of its odd extension to the period Py x Px = 2(ny-1) x 2(nx-1) up to a
// sign: for the 1-D extension y_0 = 0, y_{j+1} = x_j, y_{m+1} = 0, y_{P-1-j} = -x_j of P = 2(m+1)
// samples, Y_k = -i (S_m x)_{k-1} for k = 1..m, Y_{-k} = conj(Y_k) and Y_0 = Y_{m+1} = 0.  So
// |Y|^2 equals the squared sine coefficient, the cross products of two odd fields are the real
// products of their sine coefficients, the periodic gains are even in each wavenumber, the
// periodic update of an odd innovation stays odd, and its interior is the sine-transform update.
// The plan therefore builds the odd extensions in its own buffers (exact: copies and sign
// flips), runs the periodic analysis through the public C ABI, and copies the interior back.
//
// Layouts: user fields [F][ny][nx] row-major (x fastest), extensions [F][Py][Px]; rhat
// [n_obs][ny-2][nx-2] double extended to the periodic half spectrum [n_obs][Py][Px/2+1].

#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "../../include/fftenkf.h"

namespace fftenkf {
void set_last_error(const std::string& msg);
}

namespace {

constexpr int kThreads = 256;
constexpr int kGrid = 152 * 8;   // 8 resident CTAs on each of the 152 SMs

fftenkf_status sfail(fftenkf_status s, const std::string& msg) {
  fftenkf::set_last_error(msg);
  return s;
}

constexpr int kMaxRow = 4104;   // words of one source row in shared memory (nx <= 4097)

// dst [F][Py][Px] = odd extension of the interior of src [F][ny][nx].  One unit per source row:
// interior row sy is staged in shared memory once and written to the extension rows sy and
// Py - sy (negated), 16 bytes per store; unit sy = 0 writes the two zero rows 0 and ny - 1.
template <typename W>
__global__ void __launch_bounds__(kThreads) odd_extend_kernel(const W* __restrict__ src, W* __restrict__ dst,
                                                              int F, int ny, int nx) {
  constexpr int VEC = 16 / sizeof(W);
  const W sign = W(W(1) << (8 * sizeof(W) - 1));   // IEEE sign bit of float / bfloat16
  __shared__ W row[kMaxRow];
  const int Py = 2 * (ny - 1), Px = 2 * (nx - 1);
  const long long units = (long long)F * (ny - 1);
  for (long long u = blockIdx.x; u < units; u += gridDim.x) {
    const int f = (int)(u / (ny - 1)), sy = (int)(u % (ny - 1));
    W* d0 = dst + ((size_t)f * Py + (sy == 0 ? 0 : sy)) * Px;
    W* d1 = dst + ((size_t)f * Py + (sy == 0 ? ny - 1 : Py - sy)) * Px;
    if (sy == 0) {
      for (int v = threadIdx.x; v < Px / VEC; v += kThreads) {
        reinterpret_cast<uint4*>(d0)[v] = make_uint4(0, 0, 0, 0);
        reinterpret_cast<uint4*>(d1)[v] = make_uint4(0, 0, 0, 0);
      }
      continue;
    }
    const W* s = src + ((size_t)f * ny + sy) * nx;
    __syncthreads();   // the previous unit's readers are done with row[]
    for (int x = threadIdx.x; x < nx; x += kThreads) row[x] = s[x];
    __syncthreads();
    for (int v = threadIdx.x; v < Px / VEC; v += kThreads) {
      alignas(16) W a[VEC];
      alignas(16) W b[VEC];
#pragma unroll
      for (int i = 0; i < VEC; ++i) {
        const int x = v * VEC + i;
        W w = 0, n = 0;
        if (x >= 1 && x <= nx - 2) {
          w = row[x];
          n = W(w ^ sign);
        } else if (x >= nx) {
          n = row[Px - x];
          w = W(n ^ sign);
        }
        a[i] = w;
        b[i] = n;
      }
      reinterpret_cast<uint4*>(d0)[v] = *reinterpret_cast<const uint4*>(a);
      reinterpret_cast<uint4*>(d1)[v] = *reinterpret_cast<const uint4*>(b);
    }
  }
}

// interior of dst [F][ny][nx] = the same nodes of ext [F][Py][Px]; boundary nodes untouched.
// R rows per unit (32 KB of shared memory): the extension rows (16-byte aligned) are staged with
// 16-byte loads, all R in flight before one barrier, and each user row, whose start has any element
// alignment, is written as a scalar head up to the first 16-byte boundary, 16-byte chunks, and a
// scalar tail.
template <typename W>
__global__ void __launch_bounds__(kThreads) interior_copy_kernel(const W* __restrict__ ext, W* __restrict__ dst,
                                                                 int F, int ny, int nx) {
  constexpr int VEC = 16 / sizeof(W);
  constexpr int R = 8 / sizeof(W);   // 4 BF16 rows or 2 FP32 rows
  __shared__ __align__(16) W row[R][kMaxRow];
  const int Px = 2 * (nx - 1), Py = 2 * (ny - 1);
  const int nvec = (nx + VEC - 1) / VEC;   // vectors covering nodes [0, nx) of the row; nvec * VEC <= Px
  const int n = nx - 2;
  const long long rows = (long long)F * (ny - 2);
  const long long units = (rows + R - 1) / R;
  for (long long u = blockIdx.x; u < units; u += gridDim.x) {
    __syncthreads();   // the previous unit's readers are done with row[][]
    for (int i = threadIdx.x; i < R * nvec; i += kThreads) {
      const int rr = i / nvec, v = i - rr * nvec;
      const long long r = u * R + rr;
      if (r < rows) {
        const int f = (int)(r / (ny - 2)), y = 1 + (int)(r % (ny - 2));
        reinterpret_cast<uint4*>(row[rr])[v] =
            reinterpret_cast<const uint4*>(ext + ((size_t)f * Py + y) * Px)[v];
      }
    }
    __syncthreads();
    for (int rr = 0; rr < R; ++rr) {
      const long long r = u * R + rr;
      if (r >= rows) break;
      const int f = (int)(r / (ny - 2)), y = 1 + (int)(r % (ny - 2));
      const W* sr = row[rr];
      W* d = dst + ((size_t)f * ny + y) * nx + 1;
      const int mis = (int)(reinterpret_cast<uintptr_t>(d) % 16) / (int)sizeof(W);
      int head = (VEC - mis) % VEC;
      if (head > n) head = n;
      if ((int)threadIdx.x < head) d[threadIdx.x] = sr[1 + threadIdx.x];
      const int chunks = (n - head) / VEC;
      for (int c = threadIdx.x; c < chunks; c += kThreads) {
        alignas(16) W t[VEC];
#pragma unroll
        for (int i = 0; i < VEC; ++i) t[i] = sr[1 + head + c * VEC + i];
        reinterpret_cast<uint4*>(d + head)[c] = *reinterpret_cast<const uint4*>(t);
      }
      for (int x = head + chunks * VEC + threadIdx.x; x < n; x += kThreads) d[x] = sr[1 + x];
    }
  }
}

// periodic half-spectrum rhat [n_obs][Py][nx] (Px/2 + 1 = nx columns) from the sine rhat
// [n_obs][ny-2][nx-2]: wavenumber (k_y, k_x) takes the sine wavenumber (|k_y| - 1, k_x - 1);
// the lines where the odd extension has no content take 1 (their chat is zero, so the gain is 0)
__global__ void __launch_bounds__(kThreads) rhat_extend_kernel(const double* __restrict__ r, double* __restrict__ out,
                                                               int n_obs, int ny, int nx) {
  const int Py = 2 * (ny - 1);
  for (int row = blockIdx.x; row < n_obs * Py; row += gridDim.x) {
    const int o = row / Py, ky = row % Py;
    const int a = ky < Py - ky ? ky : Py - ky;
    const bool inside = a >= 1 && a <= ny - 2;
    const double* src = r + ((size_t)o * (ny - 2) + (inside ? a - 1 : 0)) * (nx - 2);
    double* dst = out + (size_t)row * nx;
    for (int kx = threadIdx.x; kx < nx; kx += kThreads)
      dst[kx] = (inside && kx >= 1 && kx <= nx - 2) ? src[kx - 1] : 1.0;
  }
}

// sine tables [n_auto + n_cross][ny-2][nx-2] from the periodic tables of the extension
// (n_auto real [Py][nx] tables, then n_cross complex ones, (re, im) pairs; the cross products of
// two odd fields are real, their sine product)
__global__ void __launch_bounds__(kThreads) sine_tables_kernel(const double* __restrict__ tab, double* __restrict__ out,
                                                               int n_auto, int n_cross, int ny, int nx) {
  const int my = ny - 2, mx = nx - 2, Py = 2 * (ny - 1);
  const size_t K = (size_t)Py * nx;
  const long long n = (long long)(n_auto + n_cross) * my * mx;
  for (long long i = (long long)blockIdx.x * kThreads + threadIdx.x; i < n; i += (long long)gridDim.x * kThreads) {
    const int b = (int)(i % mx);
    const int a = (int)((i / mx) % my);
    const int t = (int)(i / ((long long)mx * my));
    const size_t idx = (size_t)(a + 1) * nx + (b + 1);
    out[i] = t < n_auto ? tab[t * K + idx] : tab[n_auto * K + 2 * ((t - n_auto) * K + idx)];
  }
}

int grid_for(long long units) { return (int)(units < kGrid ? (units > 0 ? units : 1) : kGrid); }

}  // namespace

struct fftenkf_sine_plan_s {
  fftenkf_plan inner = nullptr;
  int ny, nx, Py, Px, M, N, storage, n_obs, n_un;
  size_t elem;
  void* ext_ens = nullptr;
  float* ext_data = nullptr;
  void* ext_pert = nullptr;
  double* ext_rhat = nullptr;
  double* ext_tab = nullptr;
  size_t ext_tab_doubles = 0;
};

static void release(fftenkf_sine_plan_s* p) {
  if (!p) return;
  cudaFree(p->ext_ens);
  cudaFree(p->ext_data);
  cudaFree(p->ext_pert);
  cudaFree(p->ext_rhat);
  cudaFree(p->ext_tab);
  if (p->inner) fftenkf_plan_destroy(p->inner);
  delete p;
}

static bool aligned_to(const void* q, size_t a) { return (reinterpret_cast<uintptr_t>(q) % a) == 0; }

static cudaError_t extend(const void* src, void* dst, int F, int ny, int nx, size_t elem, cudaStream_t s) {
  const long long rows = (long long)F * (ny - 1);
  if (elem == 2)
    odd_extend_kernel<uint16_t><<<grid_for(rows), kThreads, 0, s>>>(static_cast<const uint16_t*>(src),
                                                                   static_cast<uint16_t*>(dst), F, ny, nx);
  else
    odd_extend_kernel<uint32_t><<<grid_for(rows), kThreads, 0, s>>>(static_cast<const uint32_t*>(src),
                                                                   static_cast<uint32_t*>(dst), F, ny, nx);
  return cudaGetLastError();
}

extern "C" fftenkf_status fftenkf_sine_plan_create(fftenkf_sine_plan* plan, const fftenkf_dims* dims,
                                                   const uint8_t* observed_mask) {
  if (!plan || !dims || !observed_mask) return sfail(FFTENKF_EINVAL, "null argument");
  *plan = nullptr;
  const fftenkf_dims d = *dims;
  if (d.ny < 3 || d.nx < 3) return sfail(FFTENKF_EINVAL, "the grid needs interior nodes (ny, nx >= 3)");
  if (d.ny - 1 > 2048 || d.nx - 1 > 4096) return sfail(FFTENKF_EUNSUPPORTED, "ny - 1 <= 2048 and nx - 1 <= 4096");
  if ((2 * (d.nx - 1)) % 8 != 0) return sfail(FFTENKF_EUNSUPPORTED, "nx - 1 must be 2^a or 3*2^a, at least 8");
  fftenkf_dims e = d;
  e.ny = 2 * (d.ny - 1);
  e.nx = 2 * (d.nx - 1);
  fftenkf_plan inner = nullptr;
  fftenkf_status st = fftenkf_plan_create(&inner, &e, observed_mask);
  if (st != FFTENKF_OK) {
    if (st == FFTENKF_EUNSUPPORTED)
      fftenkf::set_last_error("sine plan: the odd extension 2(ny-1) x 2(nx-1) is not a supported periodic grid "
                              "(ny-1 and nx-1 must be 2^a or 3*2^a, at least 8)");
    return st;
  }
  fftenkf_sine_plan_s* p = new fftenkf_sine_plan_s();
  p->inner = inner;
  p->ny = d.ny;
  p->nx = d.nx;
  p->Py = e.ny;
  p->Px = e.nx;
  p->M = d.n_blocks;
  p->N = d.n_members;
  p->storage = d.storage;
  p->elem = d.storage == FFTENKF_BF16 ? 2 : 4;
  p->n_obs = p->n_un = 0;
  for (int j = 0; j < p->M; ++j) (observed_mask[j] ? p->n_obs : p->n_un)++;
  const size_t G = (size_t)p->Py * p->Px;
  cudaError_t ce = cudaMalloc(&p->ext_ens, (size_t)p->M * p->N * G * p->elem);
  if (ce == cudaSuccess && p->n_obs > 0) {
    ce = cudaMalloc(reinterpret_cast<void**>(&p->ext_data), (size_t)p->n_obs * G * sizeof(float));
    if (ce == cudaSuccess) ce = cudaMalloc(&p->ext_pert, (size_t)p->N * p->n_obs * G * p->elem);
    if (ce == cudaSuccess)
      ce = cudaMalloc(reinterpret_cast<void**>(&p->ext_rhat), (size_t)p->n_obs * p->Py * (p->Px / 2 + 1) * sizeof(double));
    if (ce == cudaSuccess) st = fftenkf_spectrum_size(inner, &p->ext_tab_doubles);
    if (ce == cudaSuccess && st == FFTENKF_OK)
      ce = cudaMalloc(reinterpret_cast<void**>(&p->ext_tab), p->ext_tab_doubles * sizeof(double));
  }
  if (ce != cudaSuccess) {
    release(p);
    cudaGetLastError();
    return sfail(FFTENKF_ENOMEM, std::string("sine plan buffers: ") + cudaGetErrorString(ce));
  }
  if (st != FFTENKF_OK) {
    release(p);
    return st;
  }
  *plan = p;
  return FFTENKF_OK;
}

extern "C" fftenkf_status fftenkf_sine_plan_destroy(fftenkf_sine_plan p) {
  release(p);
  return FFTENKF_OK;
}

extern "C" fftenkf_status fftenkf_sine_spectrum_size(fftenkf_sine_plan p, size_t* n_doubles) {
  if (!p || !n_doubles) return sfail(FFTENKF_EINVAL, "null argument");
  *n_doubles = (size_t)(p->n_obs + p->n_obs * p->n_un) * (p->ny - 2) * (p->nx - 2);
  return FFTENKF_OK;
}

extern "C" fftenkf_status fftenkf_sine_estimate_spectrum(fftenkf_sine_plan p, const void* ensemble,
                                                         double* spectrum_out, void* stream) {
  if (!p || !ensemble || !spectrum_out) return sfail(FFTENKF_EINVAL, "null argument");
  if (!aligned_to(ensemble, p->elem) || !aligned_to(spectrum_out, 8))
    return sfail(FFTENKF_EINVAL, "pointers must be aligned to their element type");
  if (p->n_obs == 0) return FFTENKF_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t ce = extend(ensemble, p->ext_ens, p->M * p->N, p->ny, p->nx, p->elem, s);
  if (ce != cudaSuccess) return sfail(FFTENKF_ECUDA, std::string("sine extend: ") + cudaGetErrorString(ce));
  fftenkf_status st = fftenkf_estimate_spectrum(p->inner, p->ext_ens, p->ext_tab, nullptr, stream);
  if (st != FFTENKF_OK) return st;
  const int n_cross = p->n_obs * p->n_un;
  const long long n = (long long)(p->n_obs + n_cross) * (p->ny - 2) * (p->nx - 2);
  sine_tables_kernel<<<grid_for((n + kThreads - 1) / kThreads), kThreads, 0, s>>>(p->ext_tab, spectrum_out, p->n_obs,
                                                                                 n_cross, p->ny, p->nx);
  ce = cudaGetLastError();
  if (ce != cudaSuccess) return sfail(FFTENKF_ECUDA, std::string("sine tables: ") + cudaGetErrorString(ce));
  return FFTENKF_OK;
}

extern "C" fftenkf_status fftenkf_sine_analyze(fftenkf_sine_plan p, void* ensemble, const float* data,
                                               const void* perturbations, const double* rhat, void* stream) {
  if (!p || !ensemble) return sfail(FFTENKF_EINVAL, "null argument");
  if (p->n_obs == 0) return FFTENKF_OK;   // nothing observed: the forecast is the analysis
  if (!data || !perturbations || !rhat) return sfail(FFTENKF_EINVAL, "null argument");
  if (!aligned_to(ensemble, p->elem) || !aligned_to(perturbations, p->elem) || !aligned_to(data, 4) ||
      !aligned_to(rhat, 8))
    return sfail(FFTENKF_EINVAL, "pointers must be aligned to their element type");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t ce = extend(ensemble, p->ext_ens, p->M * p->N, p->ny, p->nx, p->elem, s);
  if (ce == cudaSuccess) ce = extend(data, p->ext_data, p->n_obs, p->ny, p->nx, 4, s);
  if (ce == cudaSuccess) ce = extend(perturbations, p->ext_pert, p->N * p->n_obs, p->ny, p->nx, p->elem, s);
  if (ce == cudaSuccess) {
    rhat_extend_kernel<<<grid_for((long long)p->n_obs * p->Py), kThreads, 0, s>>>(rhat, p->ext_rhat, p->n_obs,
                                                                                 p->ny, p->nx);
    ce = cudaGetLastError();
  }
  if (ce != cudaSuccess) return sfail(FFTENKF_ECUDA, std::string("sine extend: ") + cudaGetErrorString(ce));
  fftenkf_status st = fftenkf_analyze(p->inner, p->ext_ens, p->ext_data, p->ext_pert, p->ext_rhat, nullptr, nullptr,
                                      stream);
  if (st != FFTENKF_OK) return st;
  const long long rows = (long long)p->M * p->N * (p->ny - 2);
  if (p->elem == 2)
    interior_copy_kernel<uint16_t><<<grid_for((rows + 3) / 4), kThreads, 0, s>>>(static_cast<const uint16_t*>(p->ext_ens),
                                                                      static_cast<uint16_t*>(ensemble), p->M * p->N,
                                                                      p->ny, p->nx);
  else
    interior_copy_kernel<uint32_t><<<grid_for((rows + 1) / 2), kThreads, 0, s>>>(static_cast<const uint32_t*>(p->ext_ens),
                                                                      static_cast<uint32_t*>(ensemble), p->M * p->N,
                                                                      p->ny, p->nx);
  ce = cudaGetLastError();
  if (ce != cudaSuccess) return sfail(FFTENKF_ECUDA, std::string("sine interior copy: ") + cudaGetErrorString(ce));
  return FFTENKF_OK;
}

extern "C" fftenkf_status fftenkf_sine_last_device_status(fftenkf_sine_plan p, void* stream) {
  if (!p) return sfail(FFTENKF_EINVAL, "null argument");
  return fftenkf_last_device_status(p->inner, stream);
}
