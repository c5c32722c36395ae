// Stand-alone operator-apply kernel (one launch per 1D application); the
// device code is in apply.cuh.
#include "apply.cuh"

namespace femfft {

template <int NORD, int NOUT>
__global__ void __launch_bounds__(kApplyThreads, 2) apply_kernel(ApplyParams P, int TW) {
  __shared__ ApplySmem<NORD, NOUT, kApplyThreads> S;
  apply_stage_mats<NORD, NOUT, kApplyThreads>(P, S);
  __syncthreads();
  apply_block<NORD, NOUT, kApplyThreads, true>(P, TW, blockIdx.x, S);
}

int launch_apply(const ApplyParams& P, cudaStream_t s) {
  if (P.outer * (long long)P.K * P.inner <= 0) return 0;
  int TW = 1;
  while (TW * 2 <= 32 && TW * 2 <= P.inner) TW *= 2;
  const int TE = kApplyThreads / TW;
  const long long blocks = P.outer * ((P.inner + TW - 1) / TW) * ((P.K + TE - 1) / TE);
  switch (P.n) {
#define FEMFFT_APPLY_CASE(NN)                                                              \
  case NN:                                                                                 \
    if (P.nout <= 1) apply_kernel<NN, 1><<<(unsigned)blocks, kApplyThreads, 0, s>>>(P, TW); \
    else if (P.nout <= 2) apply_kernel<NN, 2><<<(unsigned)blocks, kApplyThreads, 0, s>>>(P, TW); \
    else apply_kernel<NN, 4><<<(unsigned)blocks, kApplyThreads, 0, s>>>(P, TW);            \
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
