// Ensemble mean and the storage-independent entry points of the row passes
// (the row kernels are in k_rows.cuh).
#include "k_rows.cuh"

namespace fftenkf {

// ----------------------------------------------------------------- mean
// ubar^(j)(x) = (1/N) sum_k u_k^(j)(x).  The sum is carried as an unevaluated
// pair hi + lo with an error-free two-sum per addition, so it is exact; the mean
// is its quotient by N to within one unit in the last place (pair_div), exact
// when that quotient is a float.
__global__ void __launch_bounds__(256) mean_kernel(const MeanParams p) {
  const long long nvec = p.G / 8;
  const long long total = nvec * p.M;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(idx / nvec);
    const long long q = idx - (long long)j * nvec;
    float hi[8], lo[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) hi[e] = lo[e] = 0.f;
    // four members' loads in flight before they are summed
    for (int k0 = 0; k0 < p.N; k0 += 4) {
      float x[4][8];
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const int k = k0 + kk;
        if (k >= p.N) break;
        const size_t off = ((size_t)j * p.N + k) * (size_t)p.G + (size_t)q * 8;
        if (p.storage == kBF16) {
          const uint4 raw = __ldcs(reinterpret_cast<const uint4*>(reinterpret_cast<const __nv_bfloat16*>(p.ens) + off));
          const __nv_bfloat162* b = reinterpret_cast<const __nv_bfloat162*>(&raw);
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            float2 f = __bfloat1622float2(b[e]);
            x[kk][2 * e] = f.x;
            x[kk][2 * e + 1] = f.y;
          }
        } else {
          const float4* src = reinterpret_cast<const float4*>(reinterpret_cast<const float*>(p.ens) + off);
          float4 a = __ldcs(src), b = __ldcs(src + 1);
          x[kk][0] = a.x; x[kk][1] = a.y; x[kk][2] = a.z; x[kk][3] = a.w;
          x[kk][4] = b.x; x[kk][5] = b.y; x[kk][6] = b.z; x[kk][7] = b.w;
        }
      }
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        if (k0 + kk >= p.N) break;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const float s = hi[e] + x[kk][e];
          const float bp = s - hi[e];
          const float err = (hi[e] - (s - bp)) + (x[kk][e] - bp);
          hi[e] = s;
          lo[e] += err;
        }
      }
    }
    const float Nf = (float)p.N, inv_N = 1.0f / Nf;
    float m[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) m[e] = pair_div(hi[e], lo[e], Nf, inv_N);
    float4* dst = reinterpret_cast<float4*>(p.mean + (size_t)j * p.G + (size_t)q * 8);
    dst[0] = make_float4(m[0], m[1], m[2], m[3]);
    dst[1] = make_float4(m[4], m[5], m[6], m[7]);
  }
}

// Staged form: persistent CTAs walk chunks of P points of one block; the N members'
// chunks of the next units arrive by bulk copies (one per member) into a ring of NST
// shared-memory stages while the current unit is summed, so that up to NST N P storage
// elements per SM are in flight without holding them in registers.  Thread = P/256 consecutive points; same two-sum and quotient as mean_kernel.
template <int ST, int PPT, int NST>
__global__ void __launch_bounds__(256, 1) mean_staged_kernel(const MeanParams p) {
  constexpr int es = (ST == kBF16) ? 2 : 4;
  constexpr int P = 256 * PPT;
  extern __shared__ __align__(128) unsigned char smraw[];
  const uint32_t member_bytes = (uint32_t)P * es;
  const size_t stage_bytes = (size_t)p.N * member_bytes;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smraw + NST * stage_bytes);
  int* flag = reinterpret_cast<int*>(bars + NST);
  const long long per_block = p.G / P;
  const long long U = per_block * p.M;
  const char* ens = reinterpret_cast<const char*>(p.ens);
  auto issue = [&](long long u, int st) {
    const int j = (int)(u / per_block);
    const long long c = u - (long long)j * per_block;
    mbar_arrive_expect_tx(&bars[st], (uint32_t)stage_bytes);
    for (int k = 0; k < p.N; ++k)
      bulk_g2s(smraw + st * stage_bytes + (size_t)k * member_bytes,
               ens + (((size_t)j * p.N + k) * (size_t)p.G + (size_t)c * P) * es, member_bytes, &bars[st]);
  };
  if (threadIdx.x == 0) {
    for (int i = 0; i < NST; ++i) mbar_init(&bars[i], 1);
    mbar_fence_init();
  }
  __syncthreads();
  long long u = blockIdx.x;
  if (threadIdx.x == 0)   // units u, u + grid, ..., one per stage
    for (int i = 0; i < NST; ++i)
      if (u + (long long)i * gridDim.x < U) issue(u + (long long)i * gridDim.x, i);
  uint32_t phases = 0;   // bit i: parity to wait for on stage i
  const float Nf = (float)p.N, inv_N = 1.0f / Nf;
  for (int it = 0; u < U; u += gridDim.x, ++it) {
    const int st = it % NST;
    if (!cta_wait(&bars[st], (phases >> st) & 1u, p.status, flag)) {
      if (threadIdx.x == 0)   // copies into the other stages may still be landing
        for (int i = 1; i < NST; ++i) {
          const int o = (st + i) % NST;
          if (u + (long long)i * gridDim.x < U) mbar_wait_bounded(&bars[o], (phases >> o) & 1u);
        }
      return;
    }
    phases ^= 1u << st;
    float hi[PPT], lo[PPT];
#pragma unroll
    for (int e = 0; e < PPT; ++e) hi[e] = lo[e] = 0.f;
    const unsigned char* base = smraw + st * stage_bytes + (size_t)threadIdx.x * PPT * es;
    for (int k = 0; k < p.N; ++k) {
      float x[PPT];
      const unsigned char* src = base + (size_t)k * member_bytes;
      if constexpr (ST == kBF16) {   // PPT bfloat16 values as 8-byte words
#pragma unroll
        for (int e = 0; e < PPT; e += 4) {
          const uint2 raw = *reinterpret_cast<const uint2*>(src + 2 * e);
          const __nv_bfloat162* b = reinterpret_cast<const __nv_bfloat162*>(&raw);
          const float2 f0 = __bfloat1622float2(b[0]), f1 = __bfloat1622float2(b[1]);
          x[e] = f0.x; x[e + 1] = f0.y; x[e + 2] = f1.x; x[e + 3] = f1.y;
        }
      } else {
#pragma unroll
        for (int e = 0; e < PPT; e += 4) {
          const float4 f = *reinterpret_cast<const float4*>(src + 4 * e);
          x[e] = f.x; x[e + 1] = f.y; x[e + 2] = f.z; x[e + 3] = f.w;
        }
      }
#pragma unroll
      for (int e = 0; e < PPT; ++e) {   // error-free two-sum
        const float s = hi[e] + x[e];
        const float bp = s - hi[e];
        const float err = (hi[e] - (s - bp)) + (x[e] - bp);
        hi[e] = s;
        lo[e] += err;
      }
    }
    __syncthreads();   // stage consumed
    if (threadIdx.x == 0 && u + (long long)NST * gridDim.x < U) issue(u + (long long)NST * gridDim.x, st);
    const int j = (int)(u / per_block);
    const long long c = u - (long long)j * per_block;
    float* dst = p.mean + (size_t)j * p.G + (size_t)c * P + (size_t)threadIdx.x * PPT;
#pragma unroll
    for (int e = 0; e < PPT; e += 4)
      *reinterpret_cast<float4*>(dst + e) = make_float4(pair_div(hi[e], lo[e], Nf, inv_N), pair_div(hi[e + 1], lo[e + 1], Nf, inv_N),
                                                        pair_div(hi[e + 2], lo[e + 2], Nf, inv_N), pair_div(hi[e + 3], lo[e + 3], Nf, inv_N));
  }
}

template <int ST, int PPT, int NST>
static cudaError_t launch_mean_staged(const MeanParams& p, size_t smem, cudaStream_t s) {
  auto kern = mean_staged_kernel<ST, PPT, NST>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const long long U = (p.G / (256 * PPT)) * p.M;
  long long grid = sm_count();
  if (grid > U) grid = U;
  kern<<<(unsigned)grid, 256, smem, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_mean(const MeanParams& p, cudaStream_t s) {
  // staged form (schedule 0: 2 stages of 256 x 8 points, 1: 4 stages of 256 x 4) when the
  // chunks divide a field and the stages of the N members' chunks fit in 200 KB of shared
  // memory; otherwise the register form
  const int es = p.storage == kBF16 ? 2 : 4;
  const int ppt = p.vsel == 1 ? 4 : 8, nst = p.vsel == 1 ? 4 : 2;
  const size_t smem = (size_t)nst * p.N * 256 * ppt * es + 8 * nst + 16;
  if (p.status && p.G % (256 * ppt) == 0 && smem <= 200 * 1024) {
    if (ppt == 8)
      return p.storage == kBF16 ? launch_mean_staged<kBF16, 8, 2>(p, smem, s) : launch_mean_staged<kF32, 8, 2>(p, smem, s);
    return p.storage == kBF16 ? launch_mean_staged<kBF16, 4, 4>(p, smem, s) : launch_mean_staged<kF32, 4, 4>(p, smem, s);
  }
  const long long total = (p.G / 8) * p.M;
  long long blocks = (total + 255) / 256;
  if (blocks > 152LL * 16) blocks = 152LL * 16;
  mean_kernel<<<(int)blocks, 256, 0, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_row_fwd(const RowFwdParams& p, int n_fields, cudaStream_t s) {
  return p.storage == kBF16 ? launch_row_fwd_bf16(p, n_fields, s) : launch_row_fwd_f32(p, n_fields, s);
}

bool row_line_supported(int n) {
  switch (n) {
#define CASE(m) case m: return true;
    FFTENKF_ROW_SIZES(CASE)
#undef CASE
    default: return false;
  }
}

template <int L>
int row_inv_rows_L(int vsel, int ny, int nx, int es) {
  const int V = (vsel & 1) ? plan_V(L, 1) : plan_V(L, 0);
  RowShape s = inv_shape(L, V, ny, nx, es, (vsel & 2) != 0);
  // tensor copies need R >= 2 (16-byte rows of the box)
  return (s.R < 2 || s.smem > 227 * 1024 || s.T * s.R > 512) ? 0 : s.R;
}

int row_inv_rows(int L, int vsel, int ny, int nx, int es) {
  switch (L) {
#define CASE(n) case n: return row_inv_rows_L<n>(vsel, ny, nx, es);
    FFTENKF_ROW_SIZES(CASE)
#undef CASE
    default: return 0;
  }
}

cudaError_t launch_row_inv(const RowInvParams& p, int n_fields, cudaStream_t s) {
  return p.storage == kBF16 ? launch_row_inv_bf16(p, n_fields, s) : launch_row_inv_f32(p, n_fields, s);
}

}  // namespace fftenkf
