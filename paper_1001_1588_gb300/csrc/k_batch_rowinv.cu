// Batched inverse row pass: inverse row transforms and the in-place update.
#include "k_batch.cuh"

namespace fftenkf {

template <int L>
__device__ __forceinline__ void row_inv_dispatch(const BatchItem& it, int u, const BatchParams& p, float2* sm) {
  if (p.vsel) batch_row_inv_unit<L, plan_V(L, 1)>(it, u, p.storage, 1, sm);
  else batch_row_inv_unit<L, plan_V(L, 0)>(it, u, p.storage, 0, sm);
}

__global__ void __launch_bounds__(256) batch_row_inv_kernel(const BatchParams p) {
  extern __shared__ __align__(16) float2 bsm[];
  for (int w = blockIdx.x; w < p.n_units; w += gridDim.x) {
    const BatchUnit un = p.units[w];
    const BatchItem& it = p.items[un.item];
    switch (it.L) {
#define CASE(n) case n: row_inv_dispatch<n>(it, un.u, p, bsm); break;
      FFTENKF_BATCH_SIZES(CASE)
#undef CASE
      default: break;
    }
  }
}

cudaError_t launch_batch_row_inv(const BatchParams& p, int bt, size_t smem, int grid, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(batch_row_inv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  batch_row_inv_kernel<<<grid, bt, smem, s>>>(p);
  return cudaGetLastError();
}

}  // namespace fftenkf
