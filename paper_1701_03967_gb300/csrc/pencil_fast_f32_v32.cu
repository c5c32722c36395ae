// float32 register-radix pencil passes with 32 FFT values per thread (K >= 512),
// and the dispatch over V.
#include "pencil_fast_launch.cuh"

namespace femfft {
int launch_fast_f32_v16(int mode, int n, const FastParams& P, size_t smem, int threads, cudaStream_t s);

int launch_fast_f32(int mode, int n, const FastParams& P, size_t smem, int threads, cudaStream_t s) {
  if (P.V == 16) return launch_fast_f32_v16(mode, n, P, smem, threads, s);
  if (P.V == 32) return launch_fast_v<float, 32>(mode, n, P, smem, threads, s);
  return (int)cudaErrorInvalidValue;
}
}  // namespace femfft
