// Batched column update: forward column transform of the innovation, gain
// multiply (eq. spectral-enkf), inverse column transform.
#include "k_batch.cuh"

namespace fftenkf {

template <int NY>
__device__ __forceinline__ void col_update_dispatch_b(const BatchItem& it, int u, const BatchParams& p, float2* sm) {
  if (p.vsel) batch_col_update_unit<NY, plan_V(NY, 1)>(it, u, 1, sm);
  else batch_col_update_unit<NY, plan_V(NY, 0)>(it, u, 0, sm);
}

__global__ void __launch_bounds__(256) batch_col_update_kernel(const BatchParams p) {
  extern __shared__ __align__(16) float2 bsm[];
  for (int w = blockIdx.x; w < p.n_units; w += gridDim.x) {
    const BatchUnit un = p.units[w];
    const BatchItem& it = p.items[un.item];
    switch (it.ny) {
#define CASE(n) case n: col_update_dispatch_b<n>(it, un.u, p, bsm); break;
      FFTENKF_BATCH_SIZES(CASE)
#undef CASE
      default: break;
    }
  }
}

cudaError_t launch_batch_col_update(const BatchParams& p, int bt, size_t smem, int grid, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(batch_col_update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  batch_col_update_kernel<<<grid, bt, smem, s>>>(p);
  return cudaGetLastError();
}

}  // namespace fftenkf
