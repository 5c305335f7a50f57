// Batched passes over rows: ensemble mean, forward row transforms (anomaly or
// innovation) and inverse row transforms with the in-place update.
#include "k_batch.cuh"

namespace fftenkf {

cudaError_t launch_batch_row_inv(const BatchParams& p, int bt, size_t smem, int grid, cudaStream_t s);

__global__ void __launch_bounds__(256) batch_mean_kernel(const BatchParams p) {
  for (int w = blockIdx.x; w < p.n_units; w += gridDim.x) {
    const BatchUnit un = p.units[w];
    batch_mean_unit(p.items[un.item], un.u, p.storage);
  }
}

template <int L>
__device__ __forceinline__ void row_fwd_dispatch(const BatchItem& it, int u, const BatchParams& p, float2* sm) {
  if (p.vsel) batch_row_fwd_unit<L, plan_V(L, 1)>(it, u, p.mode, p.storage, 1, sm);
  else batch_row_fwd_unit<L, plan_V(L, 0)>(it, u, p.mode, p.storage, 0, sm);
}

__global__ void __launch_bounds__(256) batch_row_fwd_kernel(const BatchParams p) {
  extern __shared__ __align__(16) float2 bsm[];
  for (int w = blockIdx.x; w < p.n_units; w += gridDim.x) {
    const BatchUnit un = p.units[w];
    const BatchItem& it = p.items[un.item];
    switch (it.L) {
#define CASE(n) case n: row_fwd_dispatch<n>(it, un.u, p, bsm); break;
      FFTENKF_BATCH_SIZES(CASE)
#undef CASE
      default: break;
    }
  }
}

cudaError_t launch_batch_rows(int pass, const BatchParams& p, int bt, size_t smem, int grid, cudaStream_t s) {
  if (pass == kBMean) {
    batch_mean_kernel<<<grid, bt, 0, s>>>(p);
  } else if (pass == kBRowAnom || pass == kBRowInnov) {
    cudaError_t e = cudaFuncSetAttribute(batch_row_fwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    batch_row_fwd_kernel<<<grid, bt, smem, s>>>(p);
  } else {
    return launch_batch_row_inv(p, bt, smem, grid, s);
  }
  return cudaGetLastError();
}

}  // namespace fftenkf
