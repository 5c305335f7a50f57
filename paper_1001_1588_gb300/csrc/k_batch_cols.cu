// Batched column passes: spectral variance (eq. dii) per wavenumber column,
// FP64 gain chat/(chat+rhat), and the fused forward-column / gain / inverse-
// column update (eq. spectral-enkf).
#include "k_batch.cuh"

namespace fftenkf {

cudaError_t launch_batch_col_update(const BatchParams& p, int bt, size_t smem, int grid, cudaStream_t s);

template <int NY>
__device__ __forceinline__ void col_stats_dispatch_b(const BatchItem& it, int u, const BatchParams& p, float2* sm) {
  if (p.vsel) batch_col_stats_unit<NY, plan_V(NY, 1)>(it, u, 1, sm, p.status);
  else batch_col_stats_unit<NY, plan_V(NY, 0)>(it, u, 0, sm, p.status);
}

__global__ void __launch_bounds__(256) batch_col_stats_kernel(const BatchParams p) {
  extern __shared__ __align__(16) float2 bsm[];
  for (int w = blockIdx.x; w < p.n_units; w += gridDim.x) {
    const BatchUnit un = p.units[w];
    const BatchItem& it = p.items[un.item];
    switch (it.ny) {
#define CASE(n) case n: col_stats_dispatch_b<n>(it, un.u, p, bsm); break;
      FFTENKF_BATCH_SIZES(CASE)
#undef CASE
      default: break;
    }
  }
}

// FP64 gain per 32 x 32 tile of (k_x, k_y); rhat read in its [k_y][k_x] layout through shared memory
__device__ __forceinline__ double recip64_b(double x) {
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  double e = fma(-x, y, 1.0);
  y = fma(y, e, y);
  e = fma(-x, y, 1.0);
  return fma(y, e, y);
}

__global__ void __launch_bounds__(256) batch_gain_kernel(const BatchParams p) {
  __shared__ double rs[32][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8
  for (int w = blockIdx.x; w < p.n_units; w += gridDim.x) {
    const BatchUnit un = p.units[w];
    const BatchItem& it = p.items[un.item];
    const int L1 = it.L + 1;
    const int ntc = (L1 + 31) / 32;
    const int c0 = (un.u % ntc) * 32, ky0 = (un.u / ntc) * 32;
    __syncthreads();
    for (int yy = ty; yy < 32; yy += 8) {
      const int ky = ky0 + yy, c = c0 + tx;
      rs[yy][tx] = (ky < it.ny && c < L1) ? it.rhat[(size_t)ky * L1 + c] : 0.0;
    }
    __syncthreads();
    const double scale = 1.0 / ((double)it.ny * (double)it.nx);
    const int ky = ky0 + tx;
    for (int q = 0; q < 4; ++q) {
      const int cl = ty + 8 * q, c = c0 + cl;
      if (c < L1 && ky < it.ny) {
        const double a = (double)it.chat[(size_t)c * it.ny + ky];
        const double den = a + rs[tx][cl];
        double inv = (den > 1e-300) ? recip64_b(den) : ((den != 0.0) ? 1.0 / den : 0.0);
        it.gain[(size_t)c * it.ny + ky] = (float)(a * inv * scale);
      }
    }
  }
}

cudaError_t launch_batch_cols(int pass, const BatchParams& p, int bt, size_t smem, int grid, cudaStream_t s) {
  if (pass == kBStats) {
    cudaError_t e = cudaFuncSetAttribute(batch_col_stats_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    batch_col_stats_kernel<<<grid, bt, smem, s>>>(p);
  } else if (pass == kBUpdate) {
    return launch_batch_col_update(p, bt, smem, grid, s);
  } else {
    batch_gain_kernel<<<grid, 256, 0, s>>>(p);
  }
  return cudaGetLastError();
}

}  // namespace fftenkf
