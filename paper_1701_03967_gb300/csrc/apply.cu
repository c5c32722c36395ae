// Matrix-free float64 application of the FEM operators along one axis.
//
// The 1D operators calA, calC of Section 2 are sums of the element blocks A, C
// ((n+1) x (n+1), Lagrange basis on [-1, 1]) over the K elements, with the two
// boundary vertices removed; their explicit rows are the node rows and the
// interior rows of the 1D system in Section 2.  The N-D operator of Section 4
// is a sum of Kronecker products of these, so L u (and the residual
// b - L u, and the bilinear forms lam^T (dL/da_i) u) are evaluated as a short
// chain of 1D applications along the axes, e.g. in 2D
//     w = (a_1 s_1 calA_1 + c calC_1) u (axis 1), t = a_2 s_2 calA_2 u (axis 2),
//     L u = calC_2 w + calC_1 t.
// The stiffness factor of every term is applied to u itself and the mass
// factors afterwards: a stiffness applied to an intermediate that carries
// white rounding noise (such as calC_2 u) would amplify that noise by
// ~4 h^-2 |A| and floor the refinement at ~6e-9 (2D, n = 9, K = 1024).
// One thread computes the outputs of one element for all outputs of the
// launch; inputs are read through the read-only cache (along strided axes the
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

// One thread per (pencil position, element e): it produces the n outputs
// owned by element e (its interior nodes and its right vertex).  Every element
// product is evaluated in difference form, E u_e = E (u_e - u_e[0] 1) +
// u_e[0] (E 1) with the EXACT row sums E 1: the stiffness rows annihilate
// constants (Section 2, A (1..1)^T = 0), so the float64 products involve the
// differences of neighbouring nodal values instead of the values themselves,
// and the rounding of the entries of A (whose float64 row sums are ~1e-14,
// not 0) cannot act as a spurious zeroth-order term 4 h^-2 (A 1) u, which
// would shift the solution by ~6e-9 relative at K = 1024, n = 9.  For smooth u this removes
// most of the cancellation of 4 h^-2 calA u (terms ~h^-2 |u|, result ~|u|),
// which otherwise puts a rounding floor of ~1e-8 under the refined solution at
// K = 1024, n = 9.
template <int NORD, int NOUT>
__global__ void __launch_bounds__(kApplyThreads) apply_kernel(ApplyParams P) {
  constexpr int N1 = NORD + 1;
  __shared__ double mats[kApplyMaxTerms][N1 * N1];
  __shared__ double rows1[kApplyMaxTerms][N1];     // exact E (1..1)^T
  for (int t = 0; t < P.nterm; ++t) {
    for (int j = threadIdx.x; j < N1 * N1; j += blockDim.x) mats[t][j] = P.mats[t][j];
    for (int r = threadIdx.x; r < N1; r += blockDim.x) rows1[t][r] = P.rows1[t][r];
  }
  __syncthreads();

  const int K = P.K;
  const long long total = P.outer * (long long)K * P.inner;
  const long long pos = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double dotacc[kApplyMaxOut] = {0.0, 0.0, 0.0, 0.0};   // NOUT <= kApplyMaxOut
  double rr = 0.0, bb = 0.0;
  if (pos < total) {
    const long long w = pos % P.inner;
    const long long rest = pos / P.inner;
    const int e = (int)(rest % K);
    const long long o = rest / K;
    const long long line = o * (long long)P.M * P.inner + w;   // offset of index 0 of this pencil
    const bool has_node = e < K - 1;                           // right vertex is an unknown
    double acc[NOUT][NORD];
#pragma unroll
    for (int j = 0; j < NOUT; ++j)
#pragma unroll
      for (int r = 0; r < NORD; ++r) acc[j][r] = 0.0;
    for (int t = 0; t < P.nterm; ++t) {
      const double* x = P.in[P.t_src[t]];
      const double* E = mats[t];
      const double* E1 = rows1[t];
      double ue[N1], un[N1];
#pragma unroll
      for (int q = 0; q <= NORD; ++q) {
        int g = NORD * e + q - 1;
        ue[q] = (g >= 0 && g < P.M) ? __ldg(&x[line + (long long)g * P.inner]) : 0.0;
      }
      if (has_node) {
#pragma unroll
        for (int q = 0; q <= NORD; ++q) {
          int g = NORD * (e + 1) + q - 1;
          un[q] = (g < P.M) ? __ldg(&x[line + (long long)g * P.inner]) : 0.0;
        }
      }
      const double u0 = ue[0], v0 = un[0];
#pragma unroll
      for (int q = 1; q <= NORD; ++q) {
        ue[q] -= u0;
        if (has_node) un[q] -= v0;
      }
      double y[NORD];
#pragma unroll
      for (int s = 0; s < NORD - 1; ++s) {        // interior node s+1 of element e
        double v = u0 * E1[s + 1];
#pragma unroll
        for (int q = 1; q <= NORD; ++q) v = fma(E[(s + 1) * N1 + q], ue[q], v);
        y[s] = v;
      }
      if (has_node) {                              // vertex: row n of e + row 0 of e+1
        double v = u0 * E1[NORD] + v0 * E1[0];
#pragma unroll
        for (int q = 1; q <= NORD; ++q) v = fma(E[NORD * N1 + q], ue[q], v);
#pragma unroll
        for (int q = 1; q <= NORD; ++q) v = fma(E[q], un[q], v);
        y[NORD - 1] = v;
      } else {
        y[NORD - 1] = 0.0;
      }
      const int d = P.t_dst[t];
#pragma unroll
      for (int j = 0; j < NOUT; ++j)
        if (j == d)
#pragma unroll
          for (int r = 0; r < NORD; ++r) acc[j][r] += y[r];
    }
    const int nrow = has_node ? NORD : NORD - 1;
#pragma unroll
    for (int r = 0; r < NORD; ++r) {
      if (r >= nrow) break;
      const long long off = line + (long long)(NORD * e + r) * P.inner;
      if (P.dotv) {
        const double lv = __ldg(&P.dotv[off]);
#pragma unroll
        for (int j = 0; j < NOUT; ++j) dotacc[j] = fma(acc[j][r], lv, dotacc[j]);
      } else {
#pragma unroll
        for (int j = 0; j < NOUT; ++j) {
          if (j < P.nout) {
            double v = acc[j][r];
            if (j == 0 && P.addend) v += P.addend[off];
            if (j == 0 && P.base) {
              double b = __ldg(&P.base[off]);
              v = b - v;
              rr = fma(v, v, rr);
              bb = fma(b, b, bb);
            }
            if (j == 0 && P.out0_f32) P.out0_f32[off] = (float)v;
            else P.out[j][off] = v;
          }
        }
      }
    }
  }
  if (P.dotv) {
    block_accumulate<kApplyMaxOut>(dotacc, P.dots);
  } else if (P.norms) {
    double v2[2] = {rr, bb};
    block_accumulate<2>(v2, P.norms);
  }
}

int launch_apply(const ApplyParams& P, cudaStream_t s) {
  const long long total = P.outer * (long long)P.K * P.inner;
  if (total <= 0) return 0;
  const long long blocks = (total + kApplyThreads - 1) / kApplyThreads;
  switch (P.n) {
#define FEMFFT_APPLY_CASE(NN)                                                  \
  case NN:                                                                     \
    if (P.nout <= 1) apply_kernel<NN, 1><<<(unsigned)blocks, kApplyThreads, 0, s>>>(P); \
    else if (P.nout <= 2) apply_kernel<NN, 2><<<(unsigned)blocks, kApplyThreads, 0, s>>>(P); \
    else apply_kernel<NN, 4><<<(unsigned)blocks, kApplyThreads, 0, s>>>(P); \
    break;
    FEMFFT_APPLY_CASE(1) FEMFFT_APPLY_CASE(2) FEMFFT_APPLY_CASE(3) FEMFFT_APPLY_CASE(4)
    FEMFFT_APPLY_CASE(5) FEMFFT_APPLY_CASE(6) FEMFFT_APPLY_CASE(7) FEMFFT_APPLY_CASE(8)
    FEMFFT_APPLY_CASE(9)
#undef FEMFFT_APPLY_CASE
    default: return (int)cudaErrorInvalidValue;
  }
  return (int)cudaGetLastError();
}

}  // namespace femfft
