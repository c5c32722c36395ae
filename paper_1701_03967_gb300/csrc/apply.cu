// Stand-alone operator-apply kernel (one launch per 1D application); the
// device code is in apply.cuh.
#include <algorithm>

#include "../../include/femfft.h"
#include "apply.cuh"

namespace femfft {

template <int NORD, int NOUT>
__global__ void __launch_bounds__(kApplyThreads, 2) apply_kernel(ApplyParams P, int TW) {
  __shared__ ApplySmem<NORD, NOUT, kApplyThreads> S;
  apply_stage_mats<NORD, NOUT, kApplyThreads>(P, S);
  __syncthreads();
  apply_block<NORD, NOUT, kApplyThreads, true>(P, TW, blockIdx.x, S);
}

// Four resident CTAs per SM (64 registers, small spills): the kernel waits on
// latency, and 4 CTAs beat 2 (128 registers) and 3 (80) by 22 % and 7 % when
// the occupancy was chosen (2D n = 9, K = 1024 mixed step).
// LM: 1 for the lines mode of the contiguous axis, 0 otherwise (compiled
// apart so that neither pays for the other's index selects: measured 2 % on
// the 2D n = 9 headline apply)
// SUMT: two terms summed into output 0 in one set of row sums
// (elem_product_df_sum2), one accumulator; compiled for the position tiling
// only (a summed launch in lines mode takes the two-accumulator kernel).
template <int NORD, int NOUT, int LM, int SUMT>
__global__ void __launch_bounds__(kApplyThreads, 4) apply_kernel_df(ApplyParams P, int TW) {
  __shared__ ApplySmemDF<NORD, NOUT, kApplyThreads> S;
  extern __shared__ float2 tiles[];
  apply_stage_mats_df<NORD, NOUT, kApplyThreads>(P, S);
  apply_block_df<NORD, NOUT, kApplyThreads, true, LM, SUMT != 0>(P, TW, blockIdx.x, S, tiles);
}

// dynamic shared memory of a double-float launch, enabling it once per kernel
template <int NORD, int NOUT, int LM, int SUMT>
int launch_apply_df_lm(const ApplyParams& P, int TW, long long blocks, size_t smem, cudaStream_t s) {
  const int e = ensure_dyn_smem((const void*)apply_kernel_df<NORD, NOUT, LM, SUMT>, smem);
  if (e) return e;
  apply_kernel_df<NORD, NOUT, LM, SUMT><<<(unsigned)blocks, kApplyThreads, smem, s>>>(P, TW);
  return 0;
}
template <int NORD>
int launch_apply_df(const ApplyParams& P, int TW, long long blocks, size_t smem, cudaStream_t s) {
  const bool lines = P.inner == 1 && TW > 1;
  if (P.sum_terms && !lines) return launch_apply_df_lm<NORD, 1, 0, 1>(P, TW, blocks, smem, s);
  if (apply_df_nacc(P) <= 1) {
    if (lines) return launch_apply_df_lm<NORD, 1, 1, 0>(P, TW, blocks, smem, s);
    return launch_apply_df_lm<NORD, 1, 0, 0>(P, TW, blocks, smem, s);
  }
  if (lines) return launch_apply_df_lm<NORD, 2, 1, 0>(P, TW, blocks, smem, s);
  return launch_apply_df_lm<NORD, 2, 0, 0>(P, TW, blocks, smem, s);
}

int launch_apply(const ApplyParams& P, cudaStream_t s) {
  if (P.outer * (long long)P.K * P.inner <= 0) return 0;
  const int TW = apply_tile_w(P.inner, P.outer, P.K, kApplyThreads);
  const long long blocks = apply_tile_blocks(P.inner, P.outer, P.K, TW, kApplyThreads);
  if (P.df) {
    if (!apply_df_form_ok(P)) return (int)cudaErrorInvalidValue;
    int nin = 0;
    for (int i = 0; i < kApplyMaxIn; ++i) nin += P.in[i] != nullptr;
    // one tile per output at least, so that the outputs of blocks narrower
    // than a warp can leave through the tiles (coalesced) when there are more
    // outputs than inputs
    ApplyParams Pc = P;
    Pc.tile_cap = std::max(nin, P.nout);
    const size_t smem = apply_df_tile_bytes(P.n, TW, kApplyThreads, Pc.tile_cap);
    int rc = 0;
    switch (P.n) {
#define FEMFFT_APPLY_DF_CASE(NN)                                                       \
  case NN:                                                                             \
    rc = launch_apply_df<NN>(Pc, TW, blocks, smem, s);                                  \
    if (rc) return rc;                                                                 \
    break;
      FEMFFT_APPLY_DF_CASE(1) FEMFFT_APPLY_DF_CASE(2) FEMFFT_APPLY_DF_CASE(3) FEMFFT_APPLY_DF_CASE(4)
      FEMFFT_APPLY_DF_CASE(5) FEMFFT_APPLY_DF_CASE(6) FEMFFT_APPLY_DF_CASE(7) FEMFFT_APPLY_DF_CASE(8)
      FEMFFT_APPLY_DF_CASE(9)
#undef FEMFFT_APPLY_DF_CASE
      default: return (int)cudaErrorInvalidValue;
    }
    return (int)cudaGetLastError();
  }
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

extern "C" int fem_fft_apply_tiling(int64_t inner, int64_t outer, int64_t K, int* h_tw, int64_t* h_blocks) {
  if (inner < 1 || outer < 1 || K < 1 || K > (int64_t(1) << 30)) return FEM_FFT_ERR_ARG;
  const int TW = femfft::apply_tile_w(inner, outer, (int)K, femfft::kApplyThreads);
  if (h_tw) *h_tw = TW;
  if (h_blocks) *h_blocks = femfft::apply_tile_blocks(inner, outer, (int)K, TW, femfft::kApplyThreads);
  return FEM_FFT_OK;
}

extern "C" int fem_fft_apply_block_map(int64_t inner, int64_t outer, int64_t K, int64_t block, int64_t* h_o,
                                       int64_t* h_w, int64_t* h_e) {
  if (inner < 1 || outer < 1 || K < 1 || K > (int64_t(1) << 30) || !h_o || !h_w || !h_e) return FEM_FFT_ERR_ARG;
  const int TW = femfft::apply_tile_w(inner, outer, (int)K, femfft::kApplyThreads);
  if (block < 0 || block >= femfft::apply_tile_blocks(inner, outer, (int)K, TW, femfft::kApplyThreads))
    return FEM_FFT_ERR_ARG;
  const bool lines = inner == 1 && TW > 1;
  for (int t = 0; t < femfft::kApplyThreads; ++t) {
    const femfft::ApplyThread d =
        femfft::apply_decode(block, t, TW, femfft::kApplyThreads, (int)K, inner, outer, lines);
    h_o[t] = d.valid ? d.o : -1;
    h_w[t] = d.valid ? d.w : -1;
    h_e[t] = d.valid ? d.e : -1;
  }
  return FEM_FFT_OK;
}
