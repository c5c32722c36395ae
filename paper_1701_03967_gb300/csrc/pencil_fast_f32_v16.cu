// float32 register-radix pencil passes with 16 FFT values per thread (K <= 256).
#include "pencil_fast_launch.cuh"

namespace femfft {
int launch_fast_f32_v16(int mode, int n, const FastParams& P, size_t smem, int threads, cudaStream_t s) {
  return launch_fast_v<float, 16>(mode, n, P, smem, threads, s);
}
}  // namespace femfft
