// Matrix-free float64 application of the FEM operators along one axis.
//
// The 1D operators calA, calC of Section 2 are sums of the element blocks A, C
// ((n+1) x (n+1), Lagrange basis on [-1, 1]) over the K elements, with the two
// boundary vertices removed; their explicit rows are the node rows and the
// interior rows of the 1D system in Section 2.  The N-D operator of Section 4
// is a sum of Kronecker products of these, so L u (and the residual
// b - L u, and the bilinear forms lam^T (dL/da_i) u) are evaluated as a short
// chain of 1D applications along the axes, e.g. in 2D
//     t1 = calC_2 u, t2 = calA_2 u (axis 2), then
//     L u = (a_1 s_1 calA_1 + c calC_1) t1 + a_2 s_2 calC_1 t2 (axis 1).
// One thread computes one output position for all outputs of the launch;
// inputs are read through the read-only cache (along strided axes the
// threads of a warp cover consecutive positions of the contiguous axis).
#include <cuda_runtime.h>

#include "kernels.h"

namespace femfft {

constexpr int kApplyThreads = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Block sum of up to 4 values, then one atomicAdd per value.
template <int NV>
__device__ void block_accumulate(double (&v)[NV], double* dst) {
  __shared__ double red[kApplyThreads / 32][NV];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < NV; ++j) v[j] = warp_sum(v[j]);
  if (lane == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) red[wid][j] = v[j];
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      double x = lane < (int)(blockDim.x >> 5) ? red[lane][j] : 0.0;
      x = warp_sum(x);
      if (lane == 0 && x != 0.0) atomicAdd(&dst[j], x);
    }
  }
}

template <int NORD>
__global__ void __launch_bounds__(kApplyThreads) apply_kernel(ApplyParams P) {
  constexpr int N1 = NORD + 1;
  __shared__ double mats[kApplyMaxTerms][N1 * N1];
  for (int t = 0; t < P.nterm; ++t)
    for (int j = threadIdx.x; j < N1 * N1; j += blockDim.x) mats[t][j] = P.mats[t][j];
  __syncthreads();

  const long long total = P.outer * (long long)P.M * P.inner;
  const long long pos = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double acc[kApplyMaxOut] = {0.0, 0.0, 0.0, 0.0};
  double rr = 0.0, bb = 0.0;
  if (pos < total) {
    const long long w = pos % P.inner;
    const long long rest = pos / P.inner;
    const int i = (int)(rest % P.M);
    const long long o = rest / P.M;
    const long long line = o * (long long)P.M * P.inner + w;   // offset of index 0 of this pencil
    const int e = i / NORD;
    const int s = i - e * NORD;
    for (int t = 0; t < P.nterm; ++t) {
      const double* x = P.in[P.t_src[t]];
      const double* E = mats[t];
      double y = 0.0;
      // row of the element matrix for this node within element e
      const int row = (s < NORD - 1) ? s + 1 : NORD;
#pragma unroll
      for (int q = 0; q <= NORD; ++q) {
        int g = NORD * e + q - 1;
        if (g >= 0 && g < P.M) y = fma(E[row * N1 + q], __ldg(&x[line + (long long)g * P.inner]), y);
      }
      if (s == NORD - 1) {   // a vertex also belongs to element e + 1 (local node 0)
#pragma unroll
        for (int q = 0; q <= NORD; ++q) {
          int g = NORD * (e + 1) + q - 1;
          if (g < P.M) y = fma(E[q], __ldg(&x[line + (long long)g * P.inner]), y);
        }
      }
      acc[P.t_dst[t]] += y;
    }
    if (P.dotv) {
      const double lv = __ldg(&P.dotv[pos]);
#pragma unroll
      for (int j = 0; j < kApplyMaxOut; ++j) acc[j] *= lv;
    } else {
      for (int j = 0; j < P.nout; ++j) {
        double v = acc[j];
        if (j == 0 && P.base) {
          double b = __ldg(&P.base[pos]);
          v = b - v;
          rr = v * v;
          bb = b * b;
        }
        if (j == 0 && P.out0_f32) P.out0_f32[pos] = (float)v;
        else P.out[j][pos] = v;
      }
    }
  }
  if (P.dotv) {
    block_accumulate<kApplyMaxOut>(acc, P.dots);
  } else if (P.norms) {
    double v2[2] = {rr, bb};
    block_accumulate<2>(v2, P.norms);
  }
}

int launch_apply(const ApplyParams& P, cudaStream_t s) {
  const long long total = P.outer * (long long)P.M * P.inner;
  if (total <= 0) return 0;
  const long long blocks = (total + kApplyThreads - 1) / kApplyThreads;
  switch (P.n) {
#define FEMFFT_APPLY_CASE(NN) \
  case NN: apply_kernel<NN><<<(unsigned)blocks, kApplyThreads, 0, s>>>(P); break;
    FEMFFT_APPLY_CASE(1) FEMFFT_APPLY_CASE(2) FEMFFT_APPLY_CASE(3) FEMFFT_APPLY_CASE(4)
    FEMFFT_APPLY_CASE(5) FEMFFT_APPLY_CASE(6) FEMFFT_APPLY_CASE(7) FEMFFT_APPLY_CASE(8)
    FEMFFT_APPLY_CASE(9)
#undef FEMFFT_APPLY_CASE
    default: return (int)cudaErrorInvalidValue;
  }
  return (int)cudaGetLastError();
}

}  // namespace femfft
